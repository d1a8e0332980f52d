// Mixed form: operand preparation for the split-TF32 tensor-core Re->k
// contraction, and the FP32 band rotation that turns G3 into complex64 g.
//
// Real embedding of the complex product G3 = P_k G2 (Eq. 10 Fourier sum):
//   A[m][2e+t]      = (Re, Im)[t] of P_k[m][e]                       (K-major)
//   B[2j+s][2e+t]   = [[Re G2, -Im G2], [Im G2, Re G2]][s][t] at (e, j)   (K-major, one block per q)
// so that C[m][2j+s] = sum_{e,t} A[m][2e+t] B[2j+s][2e+t] is (Re, Im)[s] of G3[m][j]:
// the output is G3 as interleaved complex64.  K is zero-padded to a multiple of 32.
// Each FP64 value x is split as hi = tf32(x), lo = tf32(x - hi) (round to nearest).
#include <cuda_bf16.h>

#include "eph_kernels.cuh"

namespace eph {

__device__ __forceinline__ float tf32_rna(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

__device__ __forceinline__ void split2(double x, float& hi, float& lo) {
  hi = tf32_rna(static_cast<float>(x));
  lo = tf32_rna(static_cast<float>(x - static_cast<double>(hi)));
}

// A operand: P[n][ne] complex128 (row stride ldp) -> Ahi, Alo [n][kp] float.
__global__ void k_split_a(const double2* __restrict__ P, long ldp, int n, int ne, int kp, float* __restrict__ Ahi,
                          float* __restrict__ Alo) {
  const long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long)n * kp) return;
  const long m = idx / kp;
  const int c = (int)(idx - m * kp);
  double x = 0.0;
  if (c < 2 * ne) {
    const double2 p = P[m * ldp + (c >> 1)];
    x = (c & 1) ? p.y : p.x;
  }
  float hi, lo;
  split2(x, hi, lo);
  Ahi[idx] = hi;
  Alo[idx] = lo;
}

cudaError_t launch_split_a(const double2* P, long ldp, int n, int ne, int kp, float* Ahi, float* Alo, cudaStream_t st) {
  const long tot = (long)n * kp;
  if (tot <= 0) return cudaSuccess;
  k_split_a<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(P, ldp, n, ne, kp, Ahi, Alo), note_launch();
  return cudaGetLastError();
}

// B operand for each q of a batch: G2 = W[q][e][col0 + j] (row stride ldw, batch stride sW),
// j < ncols -> Bhi, Blo [q][2*ncols][kp].
__global__ void k_split_b(const double2* __restrict__ W, long ldw, long sW, int col0, int ncols, int ne, int kp,
                          int nq, float* __restrict__ Bhi, float* __restrict__ Blo) {
  const long per_q = 2L * ncols * kp;
  const long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= per_q * nq) return;
  const int q = (int)(idx / per_q);
  const long rem = idx - (long)q * per_q;
  const int row = (int)(rem / kp);
  const int c = (int)(rem - (long)row * kp);
  double x = 0.0;
  if (c < 2 * ne) {
    const int e = c >> 1, t = c & 1, j = row >> 1, s = row & 1;
    const double2 g = W[(long)q * sW + (long)e * ldw + col0 + j];
    // [[Re, -Im], [Im, Re]][s][t]
    x = (s == t) ? g.x : (s == 0 ? -g.y : g.y);
  }
  float hi, lo;
  split2(x, hi, lo);
  Bhi[idx] = hi;
  Blo[idx] = lo;
}

cudaError_t launch_split_b(const double2* W, long ldw, long sW, int col0, int ncols, int ne, int kp, int nq,
                           float* Bhi, float* Blo, cudaStream_t st) {
  const long tot = 2L * ncols * kp * nq;
  if (tot <= 0) return cudaSuccess;
  k_split_b<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(W, ldw, sW, col0, ncols, ne, kp, nq, Bhi, Blo), note_launch();
  return cudaGetLastError();
}

// ---- fixed-point BF16 digits (exact tensor-core accumulation) ------------------------
// x/s = sum_i d_i 2^-8(i+1) + O(2^-8n-1), integer digits |d| <= 128, digit i stored as
// d_i 2^-8i (exact in bf16); s is a power of two with |x| <= s/2 for every x of the row
// (A: all rows share sA).
// A digits: P[n][ne] complex128 (row stride ldp) -> D[ndig][n][kp] bf16 (slice stride n*kp).
__global__ void k_digits_a(const double2* __restrict__ P, long ldp, int n, int ne, int kp, double inv_s, int ndig,
                           __nv_bfloat16* __restrict__ D, long plane) {
  const long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
  const long tot = (long)n * kp;
  if (idx >= tot) return;
  const long m = idx / kp;
  const int c = (int)(idx - m * kp);
  double x = 0.0;
  if (c < 2 * ne) {
    const double2 p = P[m * ldp + (c >> 1)];
    x = (c & 1) ? p.y : p.x;
  }
  // digit i stored pre-scaled by 2^-8i (exact in bf16), so products land at their own scale
  double y = x * inv_s * 256.0, sc = 1.0;
  for (int d = 0; d < ndig; ++d) {
    const double a = rint(y);
    D[d * plane + idx] = __float2bfloat16_rn((float)(a * sc));
    y = (y - a) * 256.0;
    sc *= 0x1p-8;
  }
}

cudaError_t launch_digits_a(const double2* P, long ldp, int n, int ne, int kp, double scale, int ndig, void* D,
                            cudaStream_t st, int plane_rows) {
  const long tot = (long)n * kp;
  if (tot <= 0) return cudaSuccess;
  if (ndig < 1 || ndig > 5 || (plane_rows > 0 && plane_rows < n)) return cudaErrorInvalidValue;
  const long plane = plane_rows > 0 ? (long)plane_rows * kp : tot;
  k_digits_a<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(P, ldp, n, ne, kp, 1.0 / scale, ndig,
                                                          static_cast<__nv_bfloat16*>(D), plane), note_launch();
  return cudaGetLastError();
}

// complex64 stored as float pairs (re, im) -> complex128
__global__ void k_f32pairs_to_c128(const float2* __restrict__ X, long n, double2* __restrict__ Y) {
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float2 v = X[i];
  Y[i] = make_double2((double)v.x, (double)v.y);
}

cudaError_t launch_f32pairs_to_c128(const float2* X, long n, double2* Y, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  k_f32pairs_to_c128<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(X, n, Y), note_launch();
  return cudaGetLastError();
}

// Per output column j of each q: s = 2^(e+1) with max_e(|Re G2|, |Im G2|) = f 2^e, f in [0.5, 1).
__global__ void k_colscale_b(const double2* __restrict__ W, long ldw, long sW, int col0, int ncols, int ne, int nq,
                             float* __restrict__ sB, long nr_stride) {
  const long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long)ncols * nq) return;
  const int q = (int)(idx / ncols);
  const int j = (int)(idx - (long)q * ncols);
  double mx = 0.0;
  for (int e = 0; e < ne; ++e) {
    const double2 g = W[(long)q * sW + (long)e * ldw + col0 + j];
    mx = fmax(mx, fmax(fabs(g.x), fabs(g.y)));
  }
  float s = 1.0f;
  if (mx > 0.0) {
    int ex;
    frexp(mx, &ex);
    s = (float)ldexp(1.0, ex + 1);
  }
  sB[(long)q * nr_stride + 2 * j] = s;
  sB[(long)q * nr_stride + 2 * j + 1] = s;
}

// B digits: real embedding of columns col0.. of W (as k_split_b) scaled by sB -> D[ndig][QB*2ncols][kp].
__global__ void k_digits_b(const double2* __restrict__ W, long ldw, long sW, int col0, int ncols, int ne, int kp,
                           int nq, const float* __restrict__ sB, long slice, int ndig, __nv_bfloat16* __restrict__ D) {
  const long per_q = 2L * ncols * kp;
  const long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= per_q * nq) return;
  const int q = (int)(idx / per_q);
  const long rem = idx - (long)q * per_q;
  const int row = (int)(rem / kp);
  const int c = (int)(rem - (long)row * kp);
  double x = 0.0;
  if (c < 2 * ne) {
    const int e = c >> 1, t = c & 1, j = row >> 1, sgn = row & 1;
    const double2 g = W[(long)q * sW + (long)e * ldw + col0 + j];
    x = (sgn == t) ? g.x : (sgn == 0 ? -g.y : g.y);
  }
  // fixed point X = round(x / s 2^(8 ndig)) from the IEEE bits (integer pipe; s = 2^es), then
  // signed base-256 digits from the top, each rounded to nearest (|d| <= 128)
  const int es = (int)((__float_as_uint(sB[(long)q * 2 * ncols + row]) >> 23) & 0xFF) - 127;
  const int F = 8 * ndig;
  long long R = 0;
  {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const int e = (int)((b >> 52) & 0x7FF);
    if (e != 0) {
      const long long m = (long long)((b & 0xFFFFFFFFFFFFFULL) | (1ULL << 52));
      const int sh = (e - 1023) - 52 + F - es;  // |x / s| <= 1/2: m 2^sh < 2^(F - 1)
      if (sh >= 0)
        R = m << sh;
      else if (sh > -63)
        R = (m + (1LL << (-sh - 1))) >> (-sh);
      if (b >> 63) R = -R;
    }
  }
  float sc = 1.f;
  for (int d = 0; d < ndig - 1; ++d) {
    const int sh = 8 * (ndig - 1 - d);
    const long long a = (R + (1LL << (sh - 1))) >> sh;
    R -= a * (1LL << sh);
    D[d * slice + idx] = __float2bfloat16_rn((float)(int)a * sc);  // pre-scaled by 2^-8d, exact
    sc *= 0x1p-8f;
  }
  D[(ndig - 1) * slice + idx] = __float2bfloat16_rn((float)(int)R * sc);
}

cudaError_t launch_digits_b(const double2* W, long ldw, long sW, int col0, int ncols, int ne, int kp, int nq,
                            float* sB, void* D, long slice, int ndig, cudaStream_t st) {
  if (ndig < 1 || ndig > 5) return cudaErrorInvalidValue;
  const long cols = (long)ncols * nq;
  if (cols <= 0) return cudaSuccess;
  k_colscale_b<<<(unsigned)((cols + 255) / 256), 256, 0, st>>>(W, ldw, sW, col0, ncols, ne, nq, sB, 2L * ncols), note_launch();
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const long tot = 2L * ncols * kp * nq;
  k_digits_b<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(W, ldw, sW, col0, ncols, ne, kp, nq, sB, slice, ndig,
                                                           static_cast<__nv_bfloat16*>(D)), note_launch();
  return cudaGetLastError();
}

// H(k+q) from the float pairs of the high-precision tensor-core contraction: real outputs
// (hi, lo) at 2j (Re) and 2j + 1 (Im) -> complex128 element j, hi + lo exactly in FP64.
__global__ void k_pairs_to_c128(const float2* __restrict__ Hp, long n, double2* __restrict__ H) {
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float4 v = reinterpret_cast<const float4*>(Hp)[i];
  H[i] = make_double2((double)v.x + (double)v.y, (double)v.z + (double)v.w);
}

cudaError_t launch_pairs_to_c128(const float2* Hp, long n, double2* H, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  k_pairs_to_c128<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(Hp, n, H), note_launch();
  return cudaGetLastError();
}

// ---- band rotation with double-float accumulation ---------------------------------------
// g = V_{k+q}^H G3 V_k with G3 complex64 and V in FP64 carried as float pairs (hi + lo);
// products are formed exactly with fma and sums with two-sum, so the rotation adds no error
// beyond the final rounding of g to complex64.
namespace {
__device__ __forceinline__ float2 ff_split(double x) {
  const float h = __double2float_rn(x);
  return make_float2(h, __double2float_rn(x - (double)h));
}
// (sh, sl) += a * (bh + bl)
// __fmul_rn/__fadd_rn are never contracted into FMAs, which the error-free transforms rely on.
__device__ __forceinline__ void two_sum_acc(float& sh, float& sl, float p, float e) {
  const float s = __fadd_rn(sh, p);
  const float bb = __fsub_rn(s, sh);
  const float err = __fadd_rn(__fsub_rn(sh, __fsub_rn(s, bb)), __fsub_rn(p, bb));
  sl = __fadd_rn(sl, __fadd_rn(err, e));
  sh = s;
}
__device__ __forceinline__ void ff_mac1(float& sh, float& sl, float a, float bh, float bl) {
  const float p = __fmul_rn(a, bh);
  float e = fmaf(a, bh, -p);
  e = fmaf(a, bl, e);
  two_sum_acc(sh, sl, p, e);
}
// (sh, sl) += (ah + al) * (bh + bl)
__device__ __forceinline__ void ff_mac2(float& sh, float& sl, float ah, float al, float bh, float bl) {
  const float p = __fmul_rn(ah, bh);
  float e = fmaf(ah, bh, -p);
  e = fmaf(ah, bl, e);
  e = fmaf(al, bh, e);
  two_sum_acc(sh, sl, p, e);
}
}  // namespace

__device__ __forceinline__ float2 to_f2(float2 v) { return v; }
__device__ __forceinline__ float2 to_f2(double2 v) { return make_float2((float)v.x, (float)v.y); }

// G3 in complex64 (from the tensor-core contraction) or complex128 (from the FP64 grid path,
// rounded to complex64 on load: 6e-8 relative, as the FP32 accumulation of the former).
template <typename TIn>
__global__ void __launch_bounds__(128) k_band_rotate_ff(const TIn* __restrict__ Y, long ldy,
                                                        const double2* __restrict__ Ukq,
                                                        const double2* __restrict__ Uk, int nk, int nm, int nb,
                                                        float2* __restrict__ g, long sgq,
                                                        const int* __restrict__ keep) {
  extern __shared__ float2 smf2[];
  const int nb2 = nb * nb;
  if (keep && !keep[blockIdx.x]) {  // screened pair (uniform over the CTA): g = 0, no arithmetic
    float2* out = g + (long)(blockIdx.x / nk) * sgq + (long)(blockIdx.x % nk) * nm * nb2;
    for (int t = threadIdx.x; t < nm * nb2; t += blockDim.x) out[t] = make_float2(0.f, 0.f);
    return;
  }
  float2* ukr = smf2;            // [nb2] (hi, lo) of Re V_k
  float2* uki = ukr + nb2;       // [nb2] (hi, lo) of Im V_k
  float2* uqr = uki + nb2;
  float2* uqi = uqr + nb2;
  float2* G = uqi + nb2;         // [nm*nb2] complex64
  float2* Tr = G + nm * nb2;     // [nm*nb2] (hi, lo) of Re T
  float2* Ti = Tr + nm * nb2;    // [nm*nb2] (hi, lo) of Im T
  const long pair = blockIdx.x;
  const int k = (int)(pair % nk);
  const long q = pair / nk;
  for (int t = threadIdx.x; t < nb2; t += blockDim.x) {
    const double2 a = Uk[(long)k * nb2 + t], b = Ukq[pair * nb2 + t];
    ukr[t] = ff_split(a.x);
    uki[t] = ff_split(a.y);
    uqr[t] = ff_split(b.x);
    uqi[t] = ff_split(b.y);
  }
  const TIn* grow = Y + pair * ldy;
  for (int t = threadIdx.x; t < nm * nb2; t += blockDim.x) G[t] = to_f2(grow[t]);
  __syncthreads();
  // T[nu][a][n] = sum_b G[nu][a][b] V_k[b][n]
  for (int t = threadIdx.x; t < nm * nb2; t += blockDim.x) {
    const int nu = t / nb2, rem = t - nu * nb2, a = rem / nb, n = rem - a * nb;
    float rh = 0.f, rl = 0.f, ih = 0.f, il = 0.f;
    for (int b = 0; b < nb; ++b) {
      const float2 x = G[nu * nb2 + a * nb + b];
      const float2 ur = ukr[b * nb + n], ui = uki[b * nb + n];
      ff_mac1(rh, rl, x.x, ur.x, ur.y);
      ff_mac1(rh, rl, -x.y, ui.x, ui.y);
      ff_mac1(ih, il, x.x, ui.x, ui.y);
      ff_mac1(ih, il, x.y, ur.x, ur.y);
    }
    Tr[t] = make_float2(rh, rl);
    Ti[t] = make_float2(ih, il);
  }
  __syncthreads();
  // g[nu][m][n] = sum_a conj(V_{k+q}[a][m]) T[nu][a][n]
  float2* out = g + q * sgq + (long)k * nm * nb2;
  for (int t = threadIdx.x; t < nm * nb2; t += blockDim.x) {
    const int nu = t / nb2, rem = t - nu * nb2, m = rem / nb, n = rem - m * nb;
    float rh = 0.f, rl = 0.f, ih = 0.f, il = 0.f;
    for (int a = 0; a < nb; ++a) {
      const float2 vr = uqr[a * nb + m], vi = uqi[a * nb + m];
      const float2 tr = Tr[nu * nb2 + a * nb + n], ti = Ti[nu * nb2 + a * nb + n];
      // conj(v) t = (vr tr + vi ti) + i (vr ti - vi tr)
      ff_mac2(rh, rl, vr.x, vr.y, tr.x, tr.y);
      ff_mac2(rh, rl, vi.x, vi.y, ti.x, ti.y);
      ff_mac2(ih, il, vr.x, vr.y, ti.x, ti.y);
      ff_mac2(ih, il, -vi.x, -vi.y, tr.x, tr.y);
    }
    out[t] = make_float2(__fadd_rn(rh, rl), __fadd_rn(ih, il));
  }
}

cudaError_t launch_band_rotate_ff(const float* Y, long ldy_floats, const double2* Ukq, const double2* Uk, int nq,
                                  int nk, int nm, int nb, float* g, long sgq_floats, cudaStream_t st, const int* keep) {
  const long pairs = (long)nq * nk;
  if (pairs <= 0) return cudaSuccess;
  const size_t smem = (size_t)(4 * nb * nb + 3 * nm * nb * nb) * sizeof(float2);
  if (smem > 200 * 1024 || (ldy_floats & 1) || (sgq_floats & 1)) return cudaErrorInvalidValue;
  if (smem > 48 * 1024) {
    cudaError_t e =
        cudaFuncSetAttribute(k_band_rotate_ff<float2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  if (pairs > 2147483647L) return cudaErrorInvalidConfiguration;
  k_band_rotate_ff<float2><<<(unsigned)pairs, 128, smem, st>>>(reinterpret_cast<const float2*>(Y), ldy_floats / 2, Ukq,
                                                                Uk, nk, nm, nb, reinterpret_cast<float2*>(g),
                                                                sgq_floats / 2, keep), note_launch();
  return cudaGetLastError();
}

cudaError_t launch_band_rotate_ff_f64(const double2* Y, long ldy, const double2* Ukq, const double2* Uk, int nq, int nk,
                                      int nm, int nb, float2* g, long sgq, cudaStream_t st, const int* keep) {
  const long pairs = (long)nq * nk;
  if (pairs <= 0) return cudaSuccess;
  const size_t smem = (size_t)(4 * nb * nb + 3 * nm * nb * nb) * sizeof(float2);
  if (smem > 200 * 1024) return cudaErrorInvalidValue;
  if (smem > 48 * 1024) {
    cudaError_t e =
        cudaFuncSetAttribute(k_band_rotate_ff<double2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  if (pairs > 2147483647L) return cudaErrorInvalidConfiguration;
  k_band_rotate_ff<double2><<<(unsigned)pairs, 128, smem, st>>>(Y, ldy, Ukq, Uk, nk, nm, nb, g, sgq, keep), note_launch();
  return cudaGetLastError();
}

}  // namespace eph
